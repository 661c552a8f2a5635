"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/dmts.h declares, and its host helpers agree with
the oracle. No GPU is touched."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2602_14975_gb300 import _lib as L
from paper_2602_14975_gb300 import buildlib as B
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return L.lib()


def _declared_functions():
    hdr = open(os.path.join(ROOT, "include", "dmts.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^(?:[A-Za-z_]\w*[\s\*]+)+([A-Za-z_]\w*)\s*\(", hdr, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/dmts.h but not exported"
    assert set(declared) == set(L.EXPORTS)


def test_library_built_for_sm103a():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(L.lib_path())


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ct.c_void_p()
    st = lib.dmts_create(ct.byref(h), None, None, None, 0)
    assert st == L.E_CUDA
    assert not h.value


def test_missing_library_raises_instead_of_falling_back():
    # the product path has no CPU fallback: without the built library every
    # entry point raises (checked in a child process with the loader pointed
    # at a path that does not exist)
    import subprocess
    import sys
    code = ("import paper_2602_14975_gb300._lib as L\n"
            "L.lib_path = lambda: '/nonexistent/libdmts.so'\n"
            "try:\n    L.lib(build_if_missing=False)\nexcept RuntimeError as e:\n    print('raised', e)\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("raised"), out.stdout + out.stderr


def test_hmr_matches_oracle():
    sy = S.solvated_chain(n_chain=80, n_water=300, box_len=22.0, seed=5)
    m0 = sy.element_masses()
    a = core.masses_hmr(sy.species, sy.mol_id, m0, 3.0)
    b = O.hmr_masses(sy.species, sy.mol_id, m0, 3.0)
    assert np.abs(a - b).max() < 1e-12


def test_bond_table_lists_every_bond_twice():
    sy = S.water_192()
    ptr, idx, r0 = core.bond_table(sy.n_atoms, sy.bonds, sy.bond_r0)
    assert ptr[-1] == 2 * sy.bonds.shape[0]
    got = set()
    for i in range(sy.n_atoms):
        for q in range(ptr[i], ptr[i + 1]):
            got.add((i, int(idx[q])))
            assert abs(r0[q] - 0.9572) < 1e-6
    ref = {(int(a), int(b)) for a, b in sy.bonds} | {(int(b), int(a)) for a, b in sy.bonds}
    assert got == ref


def test_bond_table_rejects_bad_index():
    with pytest.raises(L.DmtsError):
        core.bond_table(3, np.array([[0, 5]]), np.array([1.0]))


def test_header_struct_sizes_match_ctypes(tmp_path):
    # the ctypes mirrors must have the C layout: a C program compiled against
    # include/dmts.h prints sizeof and the offset of every mirrored field
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    mirrors = {"dmts_model": L.Model, "dmts_prior": L.Prior, "dmts_system": L.System, "dmts_nbr": L.Nbr,
               "dmts_integrator": L.Integrator, "dmts_state": L.State, "dmts_request": L.Request,
               "dmts_serve_cfg": L.ServeCfg, "dmts_result": L.Result, "dmts_serve_stats": L.ServeStats,
               "dmts_guard": L.Guard, "dmts_guard_stats": L.GuardStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dmts.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ct.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
