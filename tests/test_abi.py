"""CPU checks of the C-ABI boundary: the sm_103a library builds, loads, exports
every function include/flbm.h declares, and its structs have the same layout
as the ctypes mirrors. Only host-side entry points are called here."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(flbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1909_01092_gb300 import binding
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("flbm_create", "flbm_step", "flbm_particle_state", "flbm_observables", "flbm_destroy"):
        assert must in names


def test_library_exports_every_declared_function(lib):
    from paper_1909_01092_gb300 import binding
    declared = _declared_functions()
    assert declared == set(binding.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_struct_layout_matches_ctypes(tmp_path):
    from paper_1909_01092_gb300 import binding
    src = tmp_path / "sz.c"
    src.write_text('#include "flbm.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(flbm_params), sizeof(flbm_particle),'
                   ' sizeof(flbm_obs), offsetof(flbm_params, seed), offsetof(flbm_params, pos0));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    want = [ctypes.sizeof(binding.Params), ctypes.sizeof(binding.Particle), ctypes.sizeof(binding.Obs),
            binding.Params.seed.offset, binding.Params.pos0.offset]
    assert [int(v) for v in out] == want


def test_state_bytes_and_validation(lib):
    from paper_1909_01092_gb300 import binding, workloads as W
    p = W.channel_small()
    s = binding.to_params(p)
    assert lib.flbm_state_bytes(ctypes.byref(s)) == 2 * 2 * 19 * 16 * 16 * 32 * 4
    bad = [dict(lx=0), dict(tau_s=0.5), dict(kT=-1.0), dict(wall=(2, 1, 0)), dict(init_pert=1.0),
           dict(radius=9.0), dict(radius=3.0, pos0=(1.0, 7.5, 15.5)),
           dict(radius=5.0, lz=12, wall=(1, 1, 0))]
    for over in bad:
        q = dict(p)
        q.update(over)
        assert lib.flbm_state_bytes(ctypes.byref(binding.to_params(q))) == 0, over


def test_error_strings(lib):
    for code in range(0, -7, -1):
        assert lib.flbm_error_string(code).startswith(b"FLBM_")
    assert lib.flbm_error_string(-99) == b"unknown FLBM error code"


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: if the shared object is absent, loading raises."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1909_01092_gb300 import build, binding\n"
            "build.lib_path = lambda: %r\n"
            "try:\n    binding.load(build_if_missing=False)\nexcept binding.FLBMError:\n    print('raised')\n"
            % (ROOT, str(tmp_path / "missing.so")))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert out.stdout.strip() == "raised", out.stderr
