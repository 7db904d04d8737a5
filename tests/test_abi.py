"""C-ABI checks that need no GPU: the library builds, loads and exports every
declared entry point; host-only helpers behave as documented."""
import os
import re
import ctypes as C
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "rtmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtmc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1806_00205_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for s in ("rtmc_create", "rtmc_load_mesh", "rtmc_load_see_tables", "rtmc_build_bvh", "rtmc_run"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rtmc_\w+)", out))
    missing = [s for s in _declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_loads_and_lists_exports(lib_path):
    from paper_1806_00205_gb300 import rtmc
    L = rtmc.lib()
    assert set(rtmc.EXPORTS) == set(_declared_symbols())
    for s in rtmc.EXPORTS:
        assert hasattr(L, s)


def test_binding_constants_match_the_header():
    """The binding's node formats, error codes, fates and limits are the header's #define values."""
    from paper_1806_00205_gb300 import rtmc
    src = open(os.path.join(ROOT, "include", "rtmc.h")).read()
    defs = {k: v for k, v in re.findall(r"#define\s+RTMC_(\w+)\s+\(?(-?\d+(?:\s*<<\s*\d+)?)\)?", src)}
    val = {k: eval(v) for k, v in defs.items()}          # integer literals and one shift, nothing else
    for name in ("BVH_FP32", "BVH_Q8", "BVH_W4", "BVH_Q4", "BVH_PLOC", "ESCAPED", "EMITTER", "ABSORBED_LOW",
                 "ABSORBED_OTHER", "LOST", "NOALLOC_MAX_PRIMARIES"):
        assert getattr(rtmc, name) == val[name], name
    assert rtmc.OK == val["OK"]
    for code, name in rtmc.ERRORS.items():
        assert val["ERR_" + name] == code, name


def test_record_hash_matches_documented_formula(lib_path):
    from paper_1806_00205_gb300 import rtmc
    from tests.parity import record_hashes
    rng = np.random.default_rng(0)
    rec = np.zeros(50, dtype=rtmc.RECORD_DTYPE)
    rec["prim"] = rng.integers(0, 1 << 40, 50, dtype=np.uint64)
    rec["path"] = rng.integers(1, 1 << 20, 50)
    rec["fate"] = rng.integers(0, 5, 50)
    rec["tri"] = rng.integers(-1, 10000, 50)
    rec["k"] = rng.integers(0, 16, 50)
    rec["e_bin"] = rng.integers(-1, 64, 50)
    rec["a_bin"] = rng.integers(-1, 18, 50)
    rec["wraps"] = rng.integers(0, 100, 50)
    want = record_hashes(rec)
    got = np.array([rtmc.record_hash(r) for r in rec], dtype=np.uint64)
    assert np.array_equal(got, want)


def test_create_without_gpu_fails_cleanly(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1806_00205_gb300 import rtmc
    with pytest.raises(rtmc.RtmcError):
        rtmc.Context(0)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the C struct's size and field offsets (gcc, host only)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1806_00205_gb300 import rtmc
    pairs = [("rtmc_box", rtmc.Box), ("rtmc_grid", rtmc.Grid), ("rtmc_emission", rtmc.EmissionC),
             ("rtmc_run_desc", rtmc.RunDesc), ("rtmc_batch", rtmc.Batch), ("rtmc_result", rtmc.Result),
             ("rtmc_record", rtmc.Record)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rtmc.h"', 'int main(void) {']
    for cname, py in pairs:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, py in pairs:
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
