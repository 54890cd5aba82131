"""CPU-side checks of the C ABI: the library builds, loads without a GPU,
exports every function include/crp.h declares, and the ctypes structures have
the C layout.  No compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(crp_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def crp():
    from paper_1307_2643_gb300.build import build
    build()
    from paper_1307_2643_gb300 import crp as mod
    mod.lib()
    return mod


def test_every_declared_symbol_is_exported(crp):
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(crp.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(crp.SYMBOLS) == names


def test_version_and_error_string(crp):
    assert crp.lib().crp_version() == 100
    assert isinstance(crp.lib().crp_last_error(), bytes)


def test_struct_layouts_match_c(crp, tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "crp.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(crp_grid_desc), sizeof(crp_tables_desc), sizeof(crp_candidate_arrays),"
        "sizeof(crp_modules), sizeof(crp_stats), sizeof(crp_record),"
        "offsetof(crp_modules, tables), offsetof(crp_record, status),"
        "sizeof(crp_gmf), offsetof(crp_modules, gmf), sizeof(crp_cosmology));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(crp.GridDesc), ctypes.sizeof(crp.TablesDesc),
            ctypes.sizeof(crp.CandidateArrays), ctypes.sizeof(crp.Modules),
            ctypes.sizeof(crp.Stats), crp.RECORD_DTYPE.itemsize,
            crp.Modules.tables.offset, crp.RECORD_DTYPE.fields["status"][1],
            ctypes.sizeof(crp.Gmf), crp.Modules.gmf.offset, ctypes.sizeof(crp.Cosmology)]
    assert got == want


def test_no_oracle_in_product_package():
    """The product package neither imports nor reads the oracle."""
    pkg = os.path.join(ROOT, "paper_1307_2643_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "crp_oracle" not in text and "liborc" not in text, f


def test_context_create_without_gpu_fails_cleanly(crp):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(crp.CrpError):
        crp.crp_context_create(0, 1, 16)
    assert len(crp.lib().crp_last_error()) > 0


def test_descriptors_keep_their_host_arrays_alive(crp):
    """A descriptor built from a temporary array must keep that array: the
    library copies it only later, at crp_grid_create / crp_candidates_inject."""
    import gc
    import weakref

    import numpy as np

    d = crp.grid_desc((2, 2, 2), 1.0, data=np.full((2, 2, 2, 3), 7.0))
    ref = weakref.ref(d._data_ref)
    gc.collect()
    assert ref() is not None and d.data == ref().ctypes.data
    assert float(np.ctypeslib.as_array((ctypes.c_double * 24).from_address(d.data))[5]) == 7.0

    inj = crp.host_injection(dict(x=np.arange(4.0), E=np.ones(4)))
    a = crp.candidate_arrays(inj)
    wx = weakref.ref(inj["x"])
    del inj
    gc.collect()
    assert wx() is not None and a.x == wx().ctypes.data
